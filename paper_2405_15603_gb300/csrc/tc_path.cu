// Mixed-precision path: tcgen05 BF16 tensor cores with FP32 accumulation for
// the Taylor pass, its adjoint, the weight gradient and the factor Grams;
// FP64 for the residuals, loss, factor accumulation (EMA) and everything
// downstream (inverse, preconditioning, update).
//
// Layout (per pass, per hidden layer l): activations are BF16 matrices of
// S*N_pad rows (Taylor column blocks of N_pad points, N_pad a multiple of
// 128) by hp_l = round_up(h_l, 64) features.  The value and Laplacian rows
// additionally keep the low BF16 half (x = hi + lo, split-BF16), and every
// product that produces a value or Laplacian row sums three BF16 MMAs
// (hi*hi + hi*lo + lo*hi), so the two channels the residuals depend on carry
// about 16 significant bits into the FP32 accumulator.  Tangent rows are
// plain BF16.
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include "tc_path.cuh"

#include <vector>
#include "tc_kernels.cuh"
#include "tc_engine.cuh"

using tck::Args;

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);

bool tc_make_tmap_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t stride_bytes,
                     uint32_t box_inner, uint32_t box_outer) {
    static PFN_encodeTiled_t fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = (PFN_encodeTiled_t)p;
    }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {stride_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

typedef __nv_bfloat16 bf16;
constexpr int EW = 256;
constexpr int MAX_CHUNKS = 16;
constexpr int MAX_GRAM_CHUNKS = 128;
// Longest row chunk of a Gram or weight-gradient launch: each CTA accumulates
// its chunk in FP32 (TMEM) and the chunks' partial sums are added in FP64, so
// the FP32 rounding of these sums over collocation points grows with the
// chunk, not with the whole batch (at 2048 rows it stays below the 16-bit
// split-BF16 representation error of the operands).
constexpr int GRAM_MAX_CHUNK_ROWS = 2048;

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

struct MxLayer {
    int h, hp;
    bf16 *T_hi, *T_lo, *Zb, *Gr;
    bf16 *Zb_lo, *Gr_lo;                  // split-BF16 everywhere: low halves of the adjoints
    float *A0, *AD, *SSQ, *YD;
    CUtensorMap kT_hi, kT_lo, kZb, kZb_lo;       // K-major operand maps (box 64 x 128)
    CUtensorMap gT, gZb, gGr, gT_lo, gZb_lo, gGr_lo;   // MN-major Gram maps (box 64 x 64)
};

struct MxPass {
    int N_pad, S, rows;
    MxLayer lay[KFAC_MAX_LAYERS];         // hidden layers 1..L-1 (index l-1)
    float* zl;                            // last-layer outputs, S*N_pad
    float* Xf;                            // FP32 copy of the points (N_pad x d, zero padded)
    bf16 *red_a, *red_g;                  // KFAC-reduce column sums (N_pad x hp_max)
    bf16 *red_a_lo, *red_g_lo;            // their low halves (split-BF16 everywhere)
    CUtensorMap gRa[KFAC_MAX_LAYERS], gRg[KFAC_MAX_LAYERS];
    CUtensorMap gRa_lo[KFAC_MAX_LAYERS], gRg_lo[KFAC_MAX_LAYERS];
};

struct MxWeights {
    bf16 *W_hi[KFAC_MAX_LAYERS], *W_lo[KFAC_MAX_LAYERS], *Wt[KFAC_MAX_LAYERS];
    bf16* Wt_lo[KFAC_MAX_LAYERS];         // split-BF16 everywhere: low half of Wt
    CUtensorMap kWt_lo[KFAC_MAX_LAYERS];
    float* bias[KFAC_MAX_LAYERS];
    CUtensorMap kW_hi[KFAC_MAX_LAYERS], kW_lo[KFAC_MAX_LAYERS], kWt[KFAC_MAX_LAYERS];
    CUtensorMap kWp_hi[KFAC_MAX_LAYERS], kWp_lo[KFAC_MAX_LAYERS];   // 64-row boxes (CTA pairs)
    float* wL;        // last layer weights (h_{L-1}) and bias at [hp]
    float* W1f;       // first layer in FP32, input-major: W1f[k * hp_1 + j] = W~_1[j][k], k = 0..d (d: bias)
    float* W1Qf;      // general operator: tangent inputs W_1 q_m, W1Qf[m * hp_1 + j]
};

struct MxState {
    MxPass in, bd;
    MxWeights w;
    float* part;        // tangent-chunk partials (MAX_CHUNKS x N_pad x hp_max)
    float* gpart;       // Gram partials (2 regions)
    size_t gpart_region;
    double* cs;         // column sums (4 x (hp_max + 8))
    int hp_max;
    float* Qf;          // general operator: tangent directions (d x d, FP32)
    double* gtan;       // general operator: first-layer tangent gradient sums (h_1 x d)
    float* seed;        // reverse mode: per-point seeds c_{n,s} of the interior pass (S x N_pad)
    MxWeights dw;       // KFAC*: a parameter direction converted like the weights
    bool have_dw;
    // the boundary pass runs beside the interior pass (they share only the
    // read-only weights): a stream of its own, forked from the caller's and
    // joined back
    cudaStream_t side;
    cudaEvent_t fork, join;
};

MxState* MX(kfac_pinn_handle* h) { return (MxState*)h->mx; }

template <class T>
kfac_status_t dal(T** p, size_t n) {
    void* v = nullptr;
    kfac_status_t st = kfac_device_alloc(&v, (n == 0 ? 1 : n) * sizeof(T));
    *p = (T*)v;
    return st;
}

// ============================================================================
// Element-wise kernels
// ============================================================================

// theta (FP64, column-stacked W~_l) -> BF16 hi/lo row-major W (hout_p x hin_p),
// BF16 transposed Wt (hin_p x hout_p), FP32 bias; zero padding.  One 32 x 32
// tile per block through shared memory, so that the reads (along i) and both
// layouts' writes are coalesced.
struct k_convert_weights {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ W, int hout, int hin,
                                            int hout_p, int hin_p, bf16* Whi, bf16* Wlo, bf16* Wt, bf16* Wt_lo,
                                            float* bias) {
        __shared__ float t[32][33];
        const int k0 = vb.x * 32, i0 = vb.y * 32;
        const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
        for (int kk = ty; kk < 32; kk += 8) {       // read along i
            const int i = i0 + tx, k = k0 + kk;
            // one FP64 operation per element (the conversion); the split is done in FP32
            t[kk][tx] = (i < hout && k < hin) ? (float)W[i + (long long)hout * k] : 0.f;
        }
        __syncthreads();
        for (int kk = ty; kk < 32; kk += 8) {       // W^T along i
            const int i = i0 + tx, k = k0 + kk;
            if (i >= hout_p || k >= hin_p) continue;
            const float v = t[kk][tx];
            const bf16 hi = __float2bfloat16_rn(v);
            Wt[(long long)k * hout_p + i] = hi;
            if (Wt_lo) Wt_lo[(long long)k * hout_p + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
        for (int ii = ty; ii < 32; ii += 8) {       // W along k
            const int i = i0 + ii, k = k0 + tx;
            if (i >= hout_p || k >= hin_p) continue;
            const float v = t[tx][ii];
            const bf16 hi = __float2bfloat16_rn(v);
            Whi[(long long)i * hin_p + k] = hi;
            Wlo[(long long)i * hin_p + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
        if (k0 == 0 && ty == 0 && i0 + tx < hout_p)
            bias[i0 + tx] = (i0 + tx < hout) ? (float)W[i0 + tx + (long long)hout * hin] : 0.f;
    }
};

struct k_convert_last {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ W, int hin, int hin_p, float* wL) {
        int k = vb.x * blockDim.x + threadIdx.x;
        if (k > hin_p) return;
        if (k < hin_p) wL[k] = (k < hin) ? (float)W[k] : 0.f;
        else wL[k] = (float)W[hin];     // bias at index hin_p
    }
};

// First-layer weights in FP32, input-major with the features contiguous.
struct k_convert_first {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ W, int h, int hp, int d, float* W1f) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)(d + 1) * hp) return;
        int k = (int)(idx / hp), j = (int)(idx % hp);
        W1f[idx] = (j < h) ? (float)W[j + (long long)h * k] : 0.f;
    }
};

// Points in FP32 (rows >= N zero).
struct k_points_f32 {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ X, int N, int N_pad, int d, float* Xf) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)N_pad * d) return;
        Xf[idx] = (idx < (long long)N * d) ? (float)X[idx] : 0.f;
    }
};

KFAC_DEV void store4_bf16(bf16* dst, const float* v) {
    __align__(8) __nv_bfloat162 t[2] = {__floats2bfloat162_rn(v[0], v[1]), __floats2bfloat162_rn(v[2], v[3])};
    *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(t);
}

// First layer (Sec. 3.1): inputs (x, v_1..v_d, 0), so the tangent columns of
// Z^{(1)} are W_1 v_m (Wt, input-major like W1f: the rows of W1f for v_m = e_m)
// and its Laplacian column is 0; tanh rule of Eq. 6 with channel weights chw
// (App. C.3).  FP32 arithmetic (the outputs are split-BF16, about 16 bits, at
// most); one thread per point and 4 consecutive features.
struct k_layer1 {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ W1f, const float* __restrict__ Wt,
                               const float* __restrict__ Xf, int N, int N_pad, int d, int h, int hp, int S,
                               const float* __restrict__ chw, int split_time, int split_all, bf16* T_hi, bf16* T_lo,
                               float* A0, float* AD, float* SSQ) {
        // low halves: block 0 value, 1 Laplacian, 2 time (heat); every block s at
        // its own row block when split_all
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        const int hq = hp / 4;
        if (idx >= (long long)N_pad * hq) return;
        const int n = (int)(idx / hq), j = 4 * (int)(idx % hq);
        const long long o = (long long)n * hp + j;
        const long long blk = (long long)N_pad * hp;
        float a0[4], y0[4], s1[4], hi[4], lo[4];
        bool live[4];
        {
            float4 b = *reinterpret_cast<const float4*>(W1f + (long long)d * hp + j);
            a0[0] = b.x; a0[1] = b.y; a0[2] = b.z; a0[3] = b.w;
        }
        for (int k = 0; k < d; k++) {
            const float x = Xf[(long long)n * d + k];
            float4 w = *reinterpret_cast<const float4*>(W1f + (long long)k * hp + j);
            a0[0] = fmaf(w.x, x, a0[0]); a0[1] = fmaf(w.y, x, a0[1]);
            a0[2] = fmaf(w.z, x, a0[2]); a0[3] = fmaf(w.w, x, a0[3]);
        }
        const bool row_live = n < N;
    #pragma unroll
        for (int q = 0; q < 4; q++) {
            live[q] = row_live && (j + q < h);
            a0[q] = live[q] ? a0[q] : 0.f;
            y0[q] = live[q] ? tanhf(a0[q]) : 0.f;
            s1[q] = live[q] ? 1.f - y0[q] * y0[q] : 0.f;
            __nv_bfloat16 hb = __float2bfloat16_rn(y0[q]);
            hi[q] = __bfloat162float(hb);
            lo[q] = y0[q] - hi[q];
        }
        store4_bf16(T_hi + o, hi);
        store4_bf16(T_lo + o, lo);
        float ssq[4] = {0.f, 0.f, 0.f, 0.f};
        if (S == 1) {
    #pragma unroll
            for (int q = 0; q < 4; q++) live[q] = false;   // no tangents: SSQ = 0
        }
        if (S > 1) {
            for (int i = 0; i < d; i++) {
                float4 w4 = *reinterpret_cast<const float4*>(Wt + (long long)i * hp + j);
                const float w[4] = {w4.x, w4.y, w4.z, w4.w};
                float t[4];
    #pragma unroll
                for (int q = 0; q < 4; q++) t[q] = s1[q] * w[q];
                store4_bf16(T_hi + (1 + i) * blk + o, t);
                if (split_all || (i == 0 && split_time)) {     // heat: the time tangent keeps its low half
                    float tl[4];
    #pragma unroll
                    for (int q = 0; q < 4; q++) tl[q] = t[q] - __bfloat162float(__float2bfloat16_rn(t[q]));
                    store4_bf16(T_lo + (split_all ? (1 + i) : 2) * blk + o, tl);
                }
                const float wc = chw[i];
    #pragma unroll
                for (int q = 0; q < 4; q++) ssq[q] = fmaf(wc * w[q], w[q], ssq[q]);
            }
            float dh[4], dl[4];
    #pragma unroll
            for (int q = 0; q < 4; q++) {
                if (!live[q]) ssq[q] = 0.f;
                const float yD = -2.f * y0[q] * s1[q] * ssq[q];
                __nv_bfloat16 hb = __float2bfloat16_rn(yD);
                dh[q] = __bfloat162float(hb);
                dl[q] = yD - dh[q];
            }
            store4_bf16(T_hi + (S - 1) * blk + o, dh);
            store4_bf16(T_lo + (split_all ? S - 1 : 1) * blk + o, dl);
        }
        *reinterpret_cast<float4*>(A0 + o) = make_float4(a0[0], a0[1], a0[2], a0[3]);
        *reinterpret_cast<float4*>(AD + o) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(SSQ + o) = make_float4(ssq[0], ssq[1], ssq[2], ssq[3]);
    }
};

// Laplacian row of a hidden layer once all tangent chunks are done:
// y_D = s1 a_D + s2 sum_{i in C} a_i^2  (Eq. 6).
struct k_lap_finish {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ part, int n_chunks, int N, int N_pad,
                               int h, int hp, int S, const float* __restrict__ A0, const float* __restrict__ AD,
                               float* SSQ, bf16* T_hi, bf16* T_lo, int split_all) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        const long long blk = (long long)N_pad * hp;
        if (idx >= blk) return;
        int n = (int)(idx / hp), j = (int)(idx % hp);
        float ssq = 0.f;
        for (int z = 0; z < n_chunks; z++) ssq += part[z * blk + idx];
        bool live = (n < N) && (j < h);
        float y0 = tanhf(A0[idx]);
        float s1 = 1.f - y0 * y0, s2 = -2.f * y0 * s1;
        float yD = live ? fmaf(s1, AD[idx], s2 * ssq) : 0.f;
        SSQ[idx] = live ? ssq : 0.f;
        bf16 hi = __float2bfloat16_rn(yD);
        T_hi[(S - 1) * blk + idx] = hi;
        T_lo[(split_all ? S - 1 : 1) * blk + idx] = __float2bfloat16_rn(yD - __bfloat162float(hi));
    }
};

// Last linear layer (h_L = 1): z[row] = sum_j T[row][j] w[j] (+ bias on value
// rows) for the selected Taylor blocks: all of them (nsel == 0) or the nsel
// blocks listed in sel.  One warp per row; value and Laplacian rows add their
// low halves.
struct BlockSel {
    int nsel;
    int b[3];
    int split_time;
    int split_all;      // every block has its low half at its own row block
};
struct k_last_fwd {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ T_hi, const bf16* __restrict__ T_lo,
                               const float* __restrict__ wL, int N_pad, int S, int hp, BlockSel sel, float* zl) {
        long long wid = ((long long)vb.x * blockDim.x + threadIdx.x) / 32;
        int lane = threadIdx.x % 32;
        long long nrows = (long long)(sel.nsel ? sel.nsel : S) * N_pad;
        if (wid >= nrows) return;
        int bi = (int)(wid / N_pad), n = (int)(wid % N_pad);
        int s = sel.nsel ? sel.b[bi] : bi;
        wid = (long long)s * N_pad + n;
        const bf16* row = T_hi + wid * hp;
        const bf16* lrow = nullptr;
        if (sel.split_all) lrow = T_lo + ((long long)s * N_pad + n) * hp;
        else if (s == 0) lrow = T_lo + (long long)n * hp;
        else if (s == S - 1) lrow = T_lo + ((long long)N_pad + n) * hp;
        else if (s == 1 && sel.split_time) lrow = T_lo + (2LL * N_pad + n) * hp;
        float acc = 0.f;
        for (int j = lane * 2; j < hp; j += 64) {
            float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + j));
            if (lrow) {
                float2 u = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(lrow + j));
                t.x += u.x;
                t.y += u.y;
            }
            acc = fmaf(t.x, wL[j], acc);
            acc = fmaf(t.y, wL[j + 1], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) zl[wid] = acc + (s == 0 ? wL[hp] : 0.f);
    }
};

// Residuals (Eq. 1): interior r = cT z_t + cD z_D - f, boundary r = u - g.
struct k_residual_mx {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ zl, const double* __restrict__ target,
                               double* r, int N, int N_pad, int S, int interior, double cT, double cD) {
        int n = vb.x * blockDim.x + threadIdx.x;
        if (n >= N) return;
        double v;
        if (!interior) {
            v = (double)zl[n] - target[n];
        } else {
            v = cD * (double)zl[(long long)(S - 1) * N_pad + n];
            if (cT != 0.0) v += cT * (double)zl[N_pad + n];
            v -= target[n];
        }
        r[n] = v;
    }
};

// u, grad u (rotated back to the coordinate axes when the tangent directions
// are the columns of Q) and the second-order column.
struct k_extract_mx {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ zl, int N, int N_pad, int S, int d,
                               const float* __restrict__ Qf, double* u, double* grad, double* lap) {
        int n = vb.x * blockDim.x + threadIdx.x;
        if (n >= N) return;
        if (u) u[n] = zl[n];
        if (grad) {
            for (int i = 0; i < d; i++) {
                float g;
                if (!Qf) {
                    g = zl[(long long)(1 + i) * N_pad + n];
                } else {
                    g = 0.f;
                    for (int m = 0; m < d; m++)
                        g = fmaf(Qf[(long long)i * d + m], zl[(long long)(1 + m) * N_pad + n], g);
                }
                grad[(long long)n * d + i] = g;
            }
        }
        if (lap) lap[n] = zl[(long long)(S - 1) * N_pad + n];
    }
};

// Adjoint through the last linear layer and the tanh of layer L-1: the
// incoming T^bar_s = c_s w (h_L = 1, seed c = dr/dZ^{(L)}), then the tanh
// adjoint (abar_i = s1 ybar_i - 4 y0 y_i ybar_D, ...).  Writes g = Zbar and
// r_n g for every Taylor row.
struct k_last_bwd {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ wL, const bf16* __restrict__ T_hi,
                               const float* __restrict__ A0, const float* __restrict__ AD,
                               const float* __restrict__ SSQ, const double* __restrict__ r, int N, int N_pad, int h,
                               int hp, int S, const float* __restrict__ chw, float cT, float cD,
                               const float* __restrict__ seed, bf16* Zb, bf16* Gr, const bf16* __restrict__ T_lo,
                               bf16* Zb_lo, bf16* Gr_lo) {
        // T_lo, Zb_lo, Gr_lo: split-BF16 everywhere (all three, or none)
        // seed == nullptr: the residual's constant seed c (cT, cD; 1 on the value of a
        // boundary pass); else c_{n,s} = seed[s * N_pad + n] (reverse mode of the forward
        // Laplacian).  r == nullptr: Gr = Zb.
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        const long long blk = (long long)N_pad * hp;
        if (idx >= blk) return;
        int n = (int)(idx / hp), j = (int)(idx % hp);
        bool live = (n < N) && (j < h);
        float w = live ? wL[j] : 0.f;
        float rn = (n < N) ? (r ? (float)r[n] : 1.f) : 0.f;
        float y0 = tanhf(A0[idx]);
        float s1 = 1.f - y0 * y0;
        const float c0 = seed ? seed[n] : (S == 1 ? 1.f : 0.f);
        auto put = [&](long long o, float ab) {
            const bf16 zh = __float2bfloat16_rn(ab), gh = __float2bfloat16_rn(rn * ab);
            Zb[o] = zh;
            Gr[o] = gh;
            if (Zb_lo) {
                Zb_lo[o] = __float2bfloat16_rn(ab - __bfloat162float(zh));
                Gr_lo[o] = __float2bfloat16_rn(rn * ab - __bfloat162float(gh));
            }
        };
        if (S == 1) {
            put(idx, s1 * c0 * w);
            return;
        }
        // seed c = dr/dZ^{(L)}: cD on the second-order column, cT on tangent column 1 (time, heat)
        float yD = (seed ? seed[(long long)(S - 1) * N_pad + n] : cD) * w;
        float cross = 0.f;
        for (int s = 1; s < S - 1; s++) {
            float yi = __bfloat162float(T_hi[s * blk + idx]);
            if (T_lo) yi += __bfloat162float(T_lo[s * blk + idx]);
            float ybar = (seed ? seed[(long long)s * N_pad + n] : (s == 1 ? cT : 0.f)) * w;
            float ab = s1 * ybar;
            ab -= 4.f * chw[s - 1] * y0 * yi * yD;
            cross = fmaf(yi, ybar, cross);
            ab = live ? ab : 0.f;
            put(s * blk + idx, ab);
        }
        float a0b = s1 * c0 * w - 2.f * y0 * cross - 2.f * s1 * (y0 * AD[idx] + (1.f - 3.f * y0 * y0) * SSQ[idx]) * yD;
        float aDb = s1 * yD;
        a0b = live ? a0b : 0.f;
        aDb = live ? aDb : 0.f;
        put(idx, a0b);
        put((S - 1) * blk + idx, aDb);
    }
};

// Column reductions run as 32 x 32 thread blocks: lane = column, warp = row
// group (rows strided by 32), then a deterministic sum over the 32 groups.
constexpr int RED_THREADS = 1024;
__device__ double reduce_row_groups(double v, double (*sh)[33]) {
    const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
    sh[rg][cl] = v;
    __syncthreads();
    double s = 0.0;
    if (rg == 0)
        for (int g = 0; g < 32; g++) s += sh[g][cl];
    return s;   // valid in row group 0
}

// FP64 column sums of rows [row0, row0+nrows) of a BF16 matrix (+ optional lo block).
struct k_colsum {
    static constexpr int THREADS = RED_THREADS;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ X, const bf16* __restrict__ Xlo, int hp,
                               long long row0, int nrows, int ncols, double* out) {
        __shared__ double sh[32][33];
        const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
        const int q = vb.x * 32 + cl;
        // FP32 partial sums per row group (FP64 arithmetic is scarce on this part),
        // combined in FP64
        float acc = 0.f;
        if (q < ncols)
            for (int n = rg; n < nrows; n += 32) {
                float v = __bfloat162float(X[(row0 + n) * hp + q]);
                if (Xlo) v += __bfloat162float(Xlo[(long long)n * hp + q]);
                acc += v;
            }
        double s = reduce_row_groups((double)acc, sh);
        if (rg == 0 && q < ncols) out[q] = s;
    }
};

// KFAC-reduce per-point sums over the S Taylor columns: out = scale * sum_s X_s.
// With X_lo (split-BF16 everywhere) the sum runs over hi + lo and is stored
// split again (out_lo = the rounding remainder of out).
struct k_sum_over_s {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ X, const bf16* __restrict__ X_lo,
                               int N_pad, int S, int hp, float scale, bf16* out, bf16* out_lo) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        const long long blk = (long long)N_pad * hp;
        if (idx >= blk) return;
        float acc = 0.f;
        for (int s = 0; s < S; s++) {
            acc += __bfloat162float(X[s * blk + idx]);
            if (X_lo) acc += __bfloat162float(X_lo[s * blk + idx]);
        }
        const float v = scale * acc;
        const bf16 hi = __float2bfloat16_rn(v);
        out[idx] = hi;
        if (out_lo) out_lo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
};

// Factor from Gram partials: M[p][q] = sc * sum_z part[z][min][max] (p,q < P),
// bias row/column sc_b * cs[q], corner `corner`; EMA into the FP64 factor.
struct k_factor_reduce {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ part, int nz, int P, int sym,
                               const double* cs, double sc, double sc_b, double corner, int with_bias, double* fac,
                               double beta, int* status) {
        int n = P + with_bias;
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)n * n) return;
        int p = (int)(idx / n), q = (int)(idx % n);
        double v;
        if (p < P && q < P) {
            int a = p, b = q;
            if (sym && a > b) { a = q; b = p; }
            double acc = 0.0;
            for (int z = 0; z < nz; z++) acc += (double)part[((long long)z * P + a) * P + b];
            v = sc * acc;
        } else if (p < P) {
            v = sc_b * cs[p];
        } else if (q < P) {
            v = sc_b * cs[q];
        } else {
            v = corner;
        }
        double o = beta * fac[idx] + (1.0 - beta) * v;
        if (!isfinite(o)) latch_status(status, KFAC_NONFINITE);
        fac[idx] = o;
    }
};

// Weight gradient of a layer from interior and boundary Gram partials:
// grad[i + P*q] = si * sum part_i[i][q] + sb * sum part_b[i][q] (q < Q), bias
// column q = Q from the column sums.
struct k_grad_reduce {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ pi, int zi, const float* __restrict__ pb,
                               int zb, int P, int Q, const double* csi, const double* csb, double si, double sb,
                               double* grad) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)P * (Q + 1)) return;
        int i = (int)(idx / (Q + 1)), q = (int)(idx % (Q + 1));
        double v;
        if (q < Q) {
            double a = 0.0, b = 0.0;
            for (int z = 0; z < zi; z++) a += (double)pi[((long long)z * P + i) * Q + q];
            for (int z = 0; z < zb; z++) b += (double)pb[((long long)z * P + i) * Q + q];
            v = si * a + sb * b;
        } else {
            v = si * csi[i] + sb * csb[i];
        }
        grad[i + (long long)P * q] = v;
    }
};

// First-layer input factor in closed form (Sec. 3.1: T^(0) has columns
// (x, e_1..e_d, 0) and bias row (1, 0, .., 0)).
struct k_factor_A1 {
    static constexpr int THREADS = RED_THREADS;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ X, int N, int d, int S, int reduce,
                               int boundary, double* fac, double beta, int* status) {
        __shared__ double shm[32][33];
        const int n1 = d + 1;
        const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
        const int p = vb.y, q = vb.x * 32 + cl;
        float acc = 0.f;     // FP32 partial sums per row group, combined in FP64
        const float sh = (reduce && !boundary) ? 1.f : 0.f;   // reduce: abar = (x + 1, 1) / S
        if (q < n1)
            for (int n = rg; n < N; n += 32) {
                float xp = (p < d) ? X[(long long)n * d + p] + sh : 1.f;
                float xq = (q < d) ? X[(long long)n * d + q] + sh : 1.f;
                acc = fmaf(xp, xq, acc);
            }
        double tot = reduce_row_groups((double)acc, shm);
        if (rg != 0 || q >= n1) return;
        const int idx = p * n1 + q;
        double v;
        if (boundary) v = tot / N;
        else if (reduce) v = tot / ((double)N * S * S);
        else v = (tot + ((p == q && p < d) ? (double)N : 0.0)) / ((double)N * S);
        double o = beta * fac[idx] + (1.0 - beta) * v;
        if (!isfinite(o)) latch_status(status, KFAC_NONFINITE);
        fac[idx] = o;
    }
};

// Weight gradient of the first layer:
//   (1/N) sum_n [ (r g)_{n,0} (x_n, 1)^T + sum_i (r g)_{n,i} (e_i, 0)^T ] + boundary term.
struct k_grad_layer1 {
    static constexpr int THREADS = RED_THREADS;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ Gr, const bf16* __restrict__ Grb,
                               const float* __restrict__ X, const float* __restrict__ Xb, int N, int N_pad, int Nb,
                               int d, int h, int hp, int S, double si, double sb, double* grad, double* gtan,
                               const bf16* __restrict__ Gr_lo, const bf16* __restrict__ Grb_lo) {
        // Gr_lo / Grb_lo: low halves (split-BF16 everywhere), or nullptr
        // dL/dW~_1[j][k] = si sum_n (r g_{n,0,j} x_{n,k} + sum_m r g_{n,m,j} (v_m)_k) + boundary term (sb);
        // with gtan the tangent sums t_{j,m} = si sum_n r g_{n,m,j} are written there
        // (the caller rotates them by the tangent directions), else v_m = e_m.
        __shared__ double shm[32][33];
        const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
        const int k = vb.y, j = vb.x * 32 + cl;
        const long long blk = (long long)N_pad * hp;
        float a = 0.f, t = 0.f, b = 0.f;     // FP32 partial sums per row group, combined in FP64
        if (j < h) {
            for (int n = rg; n < N; n += 32) {
                float g0 = __bfloat162float(Gr[(long long)n * hp + j]);
                if (Gr_lo) g0 += __bfloat162float(Gr_lo[(long long)n * hp + j]);
                if (k < d) {
                    a = fmaf(g0, X[(long long)n * d + k], a);
                    t += __bfloat162float(Gr[(1 + k) * blk + (long long)n * hp + j]);
                    if (Gr_lo) t += __bfloat162float(Gr_lo[(1 + k) * blk + (long long)n * hp + j]);
                } else {
                    a += g0;
                }
            }
            for (int n = rg; n < Nb; n += 32) {
                float g0 = __bfloat162float(Grb[(long long)n * hp + j]);
                if (Grb_lo) g0 += __bfloat162float(Grb_lo[(long long)n * hp + j]);
                b += (k < d) ? g0 * Xb[(long long)n * d + k] : g0;
            }
        }
        const double tv = si * (double)t;
        const double v = si * (double)a + sb * (double)b + (gtan ? 0.0 : tv);
        const double s = reduce_row_groups(v, shm);
        if (rg == 0 && j < h) grad[j + (long long)h * k] = s;
        if (gtan && k < d) {
            __syncthreads();
            const double st = reduce_row_groups(tv, shm);
            if (rg == 0 && j < h) gtan[j + (long long)h * k] = st;
        }
    }
};

// grad[j][k] += sum_m t_{j,m} (v_m)_k for the first layer's input columns k < d.
struct k_rotate_grad1 {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ gtan, const float* __restrict__ Qf,
                               int h, int d, double* grad) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)h * d) return;
        const int j = (int)(idx % h), k = (int)(idx / h);
        double acc = 0.0;
        for (int m = 0; m < d; m++) acc += gtan[j + (long long)h * m] * (double)Qf[(long long)k * d + m];
        grad[j + (long long)h * k] += acc;
    }
};

// Tangent inputs of the first layer for the directions v_m = Q e_m: W1Qf[m][j] = sum_k W1f[k][j] Q[k][m].
struct k_rotate_first {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ W1f, const float* __restrict__ Qf, int d,
                               int hp, float* W1Qf) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)d * hp) return;
        const int m = (int)(idx / hp), j = (int)(idx % hp);
        float acc = 0.f;
        for (int k = 0; k < d; k++) acc = fmaf(W1f[(long long)k * hp + j], Qf[(long long)k * d + m], acc);
        W1Qf[idx] = acc;
    }
};

// ---------------------------------------------------------------------------
// Residual Jacobian-vector products of KFAC* from the step's stored Taylor
// pass: J_n v = sum_l <dr_n / dW~_l, V~_l> with dr_n / dW~_l =
// sum_s g^{(l)}_{n,s} T^^{(l-1)T}_{n,s} (Sec. 3.2), so each layer adds
// sum_s g_{n,s}^T V~_l T^_{n,s}.  Hidden layers: the JDOT engine mode; the
// first layer (inputs (x; 1) on the value column, the tangent directions v_m
// on the tangent columns, 0 on the second-order column) and the last layer
// (h_L = 1, g = the residual seed c) below.
// ---------------------------------------------------------------------------
// First layer: jv[n] += g_{n,0}^T (V_1 x_n + b_v) + sum_m g_{n,m}^T V_1 v_m.
// V1f: the direction's first layer input-major (V1f[k * hp + j], k = d: bias);
// V1t: its tangent inputs V_1 v_m (V1t[m * hp + j]).  One block per point.
struct k_jdot_layer1 {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ V1f, const float* __restrict__ V1t,
                               const float* __restrict__ Xf, const bf16* __restrict__ G,
                               const bf16* __restrict__ G_lo, int N, int N_pad, int d, int hp, int S, double* jv) {
        __shared__ double sh[32];
        const int n = vb.x;
        const long long blk = (long long)N_pad * hp;
        float t = 0.f;
        for (int j = threadIdx.x; j < hp; j += blockDim.x) {
            float a0 = V1f[(long long)d * hp + j];
            for (int k = 0; k < d; k++) a0 = fmaf(V1f[(long long)k * hp + j], Xf[(long long)n * d + k], a0);
            const long long o = (long long)n * hp + j;
            float g0 = __bfloat162float(G[o]);
            if (G_lo) g0 += __bfloat162float(G_lo[o]);
            t = fmaf(a0, g0, t);
            if (S > 1)
                for (int m = 0; m < d; m++) {
                    float g = __bfloat162float(G[(1 + m) * blk + o]);
                    if (G_lo) g += __bfloat162float(G_lo[(1 + m) * blk + o]);
                    t = fmaf(V1t[(long long)m * hp + j], g, t);
                }
        }
        double v = t;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x % 32 == 0) sh[threadIdx.x / 32] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x / 32); w++) tot += sh[w];
            jv[n] += tot;
        }
    }
};

// jv[n] += sum over the JDOT launch's partial slots of part[slot][n].
struct k_jdot_reduce {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ part, int slots, int N, int N_pad,
                               double* jv) {
        const int n = vb.x * blockDim.x + threadIdx.x;
        if (n >= N) return;
        double acc = 0.0;
        for (int z = 0; z < slots; z++) acc += (double)part[(long long)z * N_pad + n];
        jv[n] += acc;
    }
};

struct k_residual_jvp_mx {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const float* __restrict__ jz, double* jv, int N, int N_pad, int S,
                               int interior, double cT, double cD) {
        int n = vb.x * blockDim.x + threadIdx.x;
        if (n >= N) return;
        double v;
        if (!interior) {
            v = (double)jz[n];
        } else {
            v = cD * (double)jz[(long long)(S - 1) * N_pad + n];
            if (cT != 0.0) v += cT * (double)jz[N_pad + n];
        }
        jv[n] = v;
    }
};

// Reverse mode of the forward Laplacian: the seed c_{n,s} = dphi/dZ^{(L)}_{n,s} per
// point, in FP32: the value row takes du, the tangent rows dgrad (rotated into
// the tangent directions, Q^T dgrad, for a general operator), the last row dlap.
struct k_seed_mx {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, float* seed, int N, int N_pad, int S, const float* __restrict__ Qf,
                               const double* __restrict__ du, const double* __restrict__ dgrad,
                               const double* __restrict__ dlap) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)S * N_pad) return;
        const int s = (int)(idx / N_pad), n = (int)(idx % N_pad), d = S - 2;
        float c = 0.f;
        if (n < N) {
            if (s == 0) {
                c = du ? (float)du[n] : 0.f;
            } else if (s == S - 1) {
                c = dlap ? (float)dlap[n] : 0.f;
            } else if (dgrad) {
                if (!Qf) {
                    c = (float)dgrad[(long long)n * d + (s - 1)];
                } else {
                    for (int i = 0; i < d; i++)
                        c = fmaf(Qf[(long long)i * d + (s - 1)], (float)dgrad[(long long)n * d + i], c);
                }
            }
        }
        seed[idx] = c;
    }
};

// dphi/dW~_L[q] = sum_n sum_s c_{n,s} T^_{n,s}[q]: the hidden rows with their low
// halves where they have one (value, second-order, heat time; every row at its
// own block when split_all), and the bias entry q = h_{L-1} from the value
// rows.  FP32 partial sums per row group.
struct k_last_grad_seeded {
    static constexpr int THREADS = RED_THREADS;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ T_hi, const bf16* __restrict__ T_lo,
                               const float* __restrict__ seed, int N, int N_pad, int hin, int hp, int S,
                               int split_time, int split_all, double* grad) {
        __shared__ double shm[32][33];
        const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
        const int q = vb.x * 32 + cl;
        const long long blk = (long long)N_pad * hp;
        float acc = 0.f;
        if (q < hin) {
            for (int s = 0; s < S; s++) {
                const bf16* lo = nullptr;
                if (split_all) lo = T_lo + s * blk;
                else if (s == 0) lo = T_lo;
                else if (s == S - 1) lo = T_lo + blk;
                else if (s == 1 && split_time) lo = T_lo + 2 * blk;
                for (int n = rg; n < N; n += 32) {
                    float t = __bfloat162float(T_hi[s * blk + (long long)n * hp + q]);
                    if (lo) t += __bfloat162float(lo[(long long)n * hp + q]);
                    acc = fmaf(seed[(long long)s * N_pad + n], t, acc);
                }
            }
        } else if (q == hin) {
            for (int n = rg; n < N; n += 32) acc += seed[n];
        }
        const double tot = reduce_row_groups((double)acc, shm);
        if (rg == 0 && q <= hin) grad[q] = tot;
    }
};

// dphi/dx_n = W_1^T g^{(1)}_{n,0}: x enters the value column of layer 1 only.
// Zb1_lo: the adjoint's low half (split-BF16 everywhere), or nullptr.
struct k_dX_mx {
    static constexpr int THREADS = 128;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ Zb1, const bf16* __restrict__ Zb1_lo,
                               int N, int hp, int h1, int d, const float* __restrict__ W1f, double* dX) {
        extern __shared__ float zrow[];
        const int n = vb.x;
        for (int j = threadIdx.x; j < h1; j += blockDim.x) {
            float z = __bfloat162float(Zb1[(long long)n * hp + j]);
            if (Zb1_lo) z += __bfloat162float(Zb1_lo[(long long)n * hp + j]);
            zrow[j] = z;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < d; k += blockDim.x) {
            float acc = 0.f;
            for (int j = 0; j < h1; j++) acc = fmaf(zrow[j], W1f[(long long)k * hp + j], acc);
            dX[(long long)n * d + k] = acc;
        }
    }
};

struct k_copy_or_add {
    static constexpr int THREADS = EW;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, double* dst, const double* src, long long n, int add) {
        long long i = (long long)vb.x * blockDim.x + threadIdx.x;
        if (i < n) dst[i] = add ? dst[i] + src[i] : src[i];
    }
};

// Last layer: gradient (1/N) sum_{n,s} r_n c_s T^_{n,s} + boundary, and the
// 1x1 output factors B_L.
struct k_last_layer_terms {
    static constexpr int THREADS = RED_THREADS;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const bf16* __restrict__ T_hi, const bf16* __restrict__ T_lo,
                               const bf16* __restrict__ Tb_hi, const bf16* __restrict__ Tb_lo,
                               const double* __restrict__ r, const double* __restrict__ rb, int N, int N_pad, int Nb,
                               int Nb_pad, int h, int hp, int S, double cT, double cD, int reduce, double* grad,
                               double* B_int, double* B_bdy, double beta, int* status, int split_all) {
        // low halves of the Laplacian (block 1) and time (block 2) rows, or at the
        // rows' own blocks when every row is split
        __shared__ double shm[32][33];
        const int cl = threadIdx.x % 32, rg = threadIdx.x / 32;
        const int q = vb.x * 32 + cl;
        const long long blk = (long long)N_pad * hp;
        double a = 0.0, b = 0.0;
        if (q < h) {
            for (int n = rg; n < N; n += 32) {
                double tD = (double)__bfloat162float(T_hi[(S - 1) * blk + (long long)n * hp + q]) +
                            (double)__bfloat162float(T_lo[(split_all ? S - 1 : 1) * blk + (long long)n * hp + q]);
                double v = cD * tD;
                if (cT != 0.0)     // heat: the time tangent carries its low half (block 2)
                    v += cT * ((double)__bfloat162float(T_hi[blk + (long long)n * hp + q]) +
                               (double)__bfloat162float(T_lo[(split_all ? 1 : 2) * blk + (long long)n * hp + q]));
                a += r[n] * v;
            }
            for (int n = rg; n < Nb; n += 32) {
                double t0 = (double)__bfloat162float(Tb_hi[(long long)n * hp + q]) +
                            (double)__bfloat162float(Tb_lo[(long long)n * hp + q]);
                b += rb[n] * t0;
            }
        } else if (q == h) {
            for (int n = rg; n < Nb; n += 32) b += rb[n];   // bias: c_0 = 0 in the interior
        }
        const double s = reduce_row_groups(a / N + b / Nb, shm);
        if (rg != 0 || q > h) return;
        grad[q] = s;
        if (q == 0) {
            double e = reduce ? (cD + cT) * (cD + cT) : cD * cD + cT * cT;
            double o1 = beta * B_int[0] + (1.0 - beta) * e;
            double o2 = beta * B_bdy[0] + (1.0 - beta) * 1.0;
            if (!isfinite(o1) || !isfinite(o2)) latch_status(status, KFAC_NONFINITE);
            B_int[0] = o1;
            B_bdy[0] = o2;
        }
    }
};

// ============================================================================
// Host helpers
// ============================================================================
// The engine's launch, or its record while a grouped batch step is recorded.
// pair: the CTA-pair kernel (forward modes; grid.x even).
template <int MODE, bool SPLIT>
kfac_status_t launch_engine_as(kfac_pinn_handle*, cudaStream_t s, const Args& a, dim3 grid, bool pair) {
    using C = tck::Cfg<MODE, SPLIT>;
    if (GroupRecorder* r = group_recorder()) {
        LaunchRec rec;
        rec.key = tck::engine_group_key(MODE, SPLIT, pair);
        rec.launch = tck::engine_group_launcher(MODE, SPLIT, pair);
        rec.grid = make_uint3(grid.x, grid.y, grid.z);
        rec.smem = pair ? (size_t)tck::Cfg<tck::FWD_VALUE, SPLIT, true>::SMEM : (size_t)C::SMEM;
        rec.align = (int)alignof(Args);
        rec.args.resize(sizeof(Args));
        memcpy(rec.args.data(), &a, sizeof(Args));
        rec.marker = 0;
        r->list->push_back(std::move(rec));
        return KFAC_OK;
    }
    const cudaError_t e = tck::engine_launch(MODE, SPLIT, pair, a, grid, s);
    if (e != cudaSuccess) {
        kfac_record_cuda_error(e);
        return KFAC_CUDA_ERROR;
    }
    return KFAC_OK;
}

// work: the method's FLOPs of the launch (real sizes, one product per
// contraction); exec: the tensor-core FLOPs it issues (padded tiles, every
// split-BF16 product).
template <int MODE>
kfac_status_t launch_engine(kfac_pinn_handle* h, cudaStream_t s, const Args& a, dim3 grid, int kclass, double work,
                            double exec, bool pair = false) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return KFAC_OK;
    if (group_recording())
        return a.split_all ? launch_engine_as<MODE, true>(h, s, a, grid, pair)
                           : launch_engine_as<MODE, false>(h, s, a, grid, pair);
    timer_begin(h, kclass, s);
    kfac_status_t st = a.split_all ? launch_engine_as<MODE, true>(h, s, a, grid, pair)
                                   : launch_engine_as<MODE, false>(h, s, a, grid, pair);
    if (st) return st;
    timer_end(h, kclass, s, work, exec);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

Args base_args(kfac_pinn_handle* h, const MxPass& P, int N) {
    Args a;
    memset(&a, 0, sizeof(a));
    a.N_pad = P.N_pad;
    a.N = N;
    a.S = P.S;
    a.chw = h->chw32;
    a.split_time = (h->cfg.op == KFAC_OP_HEAT && P.S > 2) ? 1 : 0;
    a.split_all = is_split_all(h) ? 1 : 0;
    a.status = h->status;
    return a;
}

// Fraction of the SM-time of ceil(ctas / sm) full waves that `ctas` equal CTAs
// (one per SM at a time) keep busy.
double wave_efficiency(long long ctas, int sm) {
    const long long waves = (ctas + sm - 1) / sm;
    return (double)ctas / (double)(waves * sm);
}

// Candidate chunk lengths of one split-K launch with the wave model's
// efficiency (the fraction of full waves kept busy times the fraction of
// chunk slots holding work); `model` is the first of the highest efficiency,
// so ties keep fewer, longer chunks (fewer partial sums to combine).
struct Cands {
    int n = 0, model = 0;
    int len[64];
    double eff[64];
    void add(int c, double e) {
        for (int i = 0; i < n; i++)
            if (len[i] == c) return;
        if (n == 64) return;
        len[n] = c;
        eff[n] = e;
        if (e > eff[model] + 1e-9) model = n;
        n++;
    }
};

// Chunks of the S_tiles tangent tiles of each of `blocks` output tiles, one
// CTA per (output tile, chunk), at most MAX_CHUNKS chunks.
Cands tangent_candidates(int S_tiles, int blocks, int sm) {
    Cands c;
    const int top = S_tiles < MAX_CHUNKS ? S_tiles : MAX_CHUNKS;
    for (int n = 1; n <= top; n++) {
        const int len = (S_tiles + n - 1) / n;
        const int cnt = (S_tiles + len - 1) / len;
        c.add(len, wave_efficiency((long long)blocks * cnt, sm) * (double)S_tiles / ((double)cnt * len));
    }
    return c;
}

void choose_chunks(int S_tiles, int blocks, int sm, int& chunk_len, int& n_chunks) {
    const Cands c = tangent_candidates(S_tiles, blocks, sm);
    chunk_len = c.len[c.model];
    n_chunks = (S_tiles + chunk_len - 1) / chunk_len;
}

// ------------------------------------------------------- split-K autotuner
// The handle's table maps a launch shape to a chunk length (see
// kfac_pinn_set_autotune).  With autotuning enabled and the stream not
// capturing, an unseen shape is timed at the model's length and up to three
// runners-up by the model (one warm-up and TUNE_REPS timed launches each);
// the fastest is recorded.  Every candidate is a length the model could
// pick, so it fits the partial-sum workspace.
constexpr int TUNE_CANDIDATES = 4;
constexpr int TUNE_REPS = 3;

bool same_shape(const kfac_tune_entry_t& a, const kfac_tune_entry_t& b) {
    return a.kind == b.kind && a.P == b.P && a.Q == b.Q && a.K == b.K && a.tiles == b.tiles && a.sym == b.sym &&
           a.split == b.split;
}

int tune_find(const kfac_pinn_handle* h, const kfac_tune_entry_t& key) {
    for (int i = 0; i < h->n_tune; i++)
        if (same_shape(h->tune[i], key)) return i;
    return -1;
}

bool tune_may_measure(const kfac_pinn_handle* h, cudaStream_t s) {
    if (!h->autotune || h->n_tune >= KFAC_TUNE_CAP || group_recording()) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

// Time launch(len) over the candidates, record the fastest in the table and
// return it in `best`.  The caller launches once more with `best`.
template <class F>
kfac_status_t tune_measure(kfac_pinn_handle* h, cudaStream_t s, kfac_tune_entry_t key, const Cands& c, F&& launch,
                           int& best) {
    int order[TUNE_CANDIDATES];
    int no = 0;
    order[no++] = c.model;
    while (no < TUNE_CANDIDATES && no < c.n) {
        int pick = -1;
        for (int i = 0; i < c.n; i++) {
            bool used = false;
            for (int j = 0; j < no; j++) used = used || order[j] == i;
            if (!used && (pick < 0 || c.eff[i] > c.eff[pick] + 1e-9)) pick = i;
        }
        order[no++] = pick;
    }
    for (cudaEvent_t& e : h->tune_ev)
        if (!e) KFAC_CUDA_TRY(cudaEventCreate(&e));
    float t_best = 0.f, t_model = 0.f;
    best = c.len[c.model];
    for (int k = 0; k < no; k++) {
        const int len = c.len[order[k]];
        kfac_status_t st = launch(len);   // warm-up
        if (st) return st;
        KFAC_CUDA_TRY(cudaEventRecord(h->tune_ev[0], s));
        for (int r = 0; r < TUNE_REPS; r++)
            if ((st = launch(len))) return st;
        KFAC_CUDA_TRY(cudaEventRecord(h->tune_ev[1], s));
        KFAC_CUDA_TRY(cudaEventSynchronize(h->tune_ev[1]));
        float ms = 0.f;
        KFAC_CUDA_TRY(cudaEventElapsedTime(&ms, h->tune_ev[0], h->tune_ev[1]));
        const float us = 1000.f * ms / TUNE_REPS;
        if (k == 0) t_model = us;
        if (k == 0 || us < t_best) {
            t_best = us;
            best = len;
        }
    }
    key.chunk = best;
    key.model_chunk = c.len[c.model];
    key.us = t_best;
    key.model_us = t_model;
    h->tune[h->n_tune++] = key;
    return KFAC_OK;
}

// Tangent-tile chunk length of a FWD_TAN / BWD_TAN launch: the table's, else
// the model's, measured first when the tuner may.
template <class F>
kfac_status_t tangent_chunk(kfac_pinn_handle* h, cudaStream_t s, int kind, int split, int N_pad, int hp_out,
                            int hp_in, int S_tiles, int blocks, F&& launch, int& len) {
    const Cands c = tangent_candidates(S_tiles, blocks, h->sm_count);
    len = c.len[c.model];
    kfac_tune_entry_t key;
    memset(&key, 0, sizeof(key));
    key.kind = kind;
    key.P = N_pad;
    key.Q = hp_out;
    key.K = hp_in;
    key.tiles = S_tiles;
    key.split = split;
    const int ti = tune_find(h, key);
    if (ti >= 0) {
        const int t = h->tune[ti].chunk;
        if (t >= 1 && t <= S_tiles && (S_tiles + t - 1) / t <= MAX_CHUNKS) len = t;
        return KFAC_OK;
    }
    if (tune_may_measure(h, s)) return tune_measure(h, s, key, c, launch, len);
    return KFAC_OK;
}

kfac_status_t alloc_pass(kfac_pinn_handle* h, MxPass& P, int Nmax, int S) {
    const int L = h->cfg.L;
    P.N_pad = round_up(Nmax, 128);
    P.S = S;
    P.rows = S * P.N_pad;
    kfac_status_t st;
    int hp_max = 64;
    for (int l = 1; l <= L - 1; l++) {
        MxLayer& ly = P.lay[l - 1];
        ly.h = h->dims[l];
        ly.hp = round_up(ly.h, 64);
        if (ly.hp > hp_max) hp_max = ly.hp;
        size_t big = (size_t)P.rows * ly.hp, small = (size_t)P.N_pad * ly.hp;
        // low halves: the value, Laplacian and (heat) time blocks, or every
        // block (laid out like the high halves) when every row is split
        const bool sa = is_split_all(h);
        const size_t lo_rows = sa ? (size_t)P.rows : 3 * (size_t)P.N_pad;
        if ((st = dal(&ly.T_hi, big))) return st;
        if ((st = dal(&ly.T_lo, lo_rows * ly.hp))) return st;
        if ((st = dal(&ly.Zb, big))) return st;
        if ((st = dal(&ly.Gr, big))) return st;
        if (sa) {
            if ((st = dal(&ly.Zb_lo, big))) return st;
            if ((st = dal(&ly.Gr_lo, big))) return st;
            cudaMemset(ly.Zb_lo, 0, big * sizeof(bf16));
            cudaMemset(ly.Gr_lo, 0, big * sizeof(bf16));
            bool ok = tc_make_tmap_2d(&ly.kZb_lo, ly.Zb_lo, ly.hp, P.rows, ly.hp * 2, 64, 128) &&
                      tc_make_tmap_2d(&ly.gT_lo, ly.T_lo, ly.hp, P.rows, ly.hp * 2, 64, 64) &&
                      tc_make_tmap_2d(&ly.gZb_lo, ly.Zb_lo, ly.hp, P.rows, ly.hp * 2, 64, 64) &&
                      tc_make_tmap_2d(&ly.gGr_lo, ly.Gr_lo, ly.hp, P.rows, ly.hp * 2, 64, 64);
            if (!ok) return KFAC_CUDA_ERROR;
        }
        if ((st = dal(&ly.A0, small))) return st;
        if ((st = dal(&ly.AD, small))) return st;
        if ((st = dal(&ly.SSQ, small))) return st;
        if ((st = dal(&ly.YD, small))) return st;
        cudaMemset(ly.T_hi, 0, big * sizeof(bf16));
        cudaMemset(ly.T_lo, 0, lo_rows * ly.hp * sizeof(bf16));
        cudaMemset(ly.Zb, 0, big * sizeof(bf16));
        cudaMemset(ly.Gr, 0, big * sizeof(bf16));
        bool ok = tc_make_tmap_2d(&ly.kT_hi, ly.T_hi, ly.hp, P.rows, ly.hp * 2, 64, 128) &&
                  tc_make_tmap_2d(&ly.kT_lo, ly.T_lo, ly.hp, lo_rows, ly.hp * 2, 64, 128) &&
                  tc_make_tmap_2d(&ly.kZb, ly.Zb, ly.hp, P.rows, ly.hp * 2, 64, 128) &&
                  tc_make_tmap_2d(&ly.gT, ly.T_hi, ly.hp, P.rows, ly.hp * 2, 64, 64) &&
                  tc_make_tmap_2d(&ly.gZb, ly.Zb, ly.hp, P.rows, ly.hp * 2, 64, 64) &&
                  tc_make_tmap_2d(&ly.gGr, ly.Gr, ly.hp, P.rows, ly.hp * 2, 64, 64);
        if (!ok) return KFAC_CUDA_ERROR;
    }
    if ((st = dal(&P.zl, (size_t)P.rows))) return st;
    if ((st = dal(&P.Xf, (size_t)P.N_pad * h->dims[0]))) return st;
    if (S > 1 && h->cfg.variant == KFAC_REDUCE) {
        const bool sa = is_split_all(h);
        if ((st = dal(&P.red_a, (size_t)P.N_pad * hp_max))) return st;
        if ((st = dal(&P.red_g, (size_t)P.N_pad * hp_max))) return st;
        if (sa) {
            if ((st = dal(&P.red_a_lo, (size_t)P.N_pad * hp_max))) return st;
            if ((st = dal(&P.red_g_lo, (size_t)P.N_pad * hp_max))) return st;
        }
        for (int l = 1; l <= L - 1; l++) {
            int hp = P.lay[l - 1].hp;
            if (!tc_make_tmap_2d(&P.gRa[l - 1], P.red_a, hp, P.N_pad, hp * 2, 64, 64) ||
                !tc_make_tmap_2d(&P.gRg[l - 1], P.red_g, hp, P.N_pad, hp * 2, 64, 64))
                return KFAC_CUDA_ERROR;
            if (sa && (!tc_make_tmap_2d(&P.gRa_lo[l - 1], P.red_a_lo, hp, P.N_pad, hp * 2, 64, 64) ||
                       !tc_make_tmap_2d(&P.gRg_lo[l - 1], P.red_g_lo, hp, P.N_pad, hp * 2, 64, 64)))
                return KFAC_CUDA_ERROR;
        }
    }
    return KFAC_OK;
}

void free_pass(MxPass& P) {
    for (int l = 0; l < KFAC_MAX_LAYERS; l++) {
        MxLayer& ly = P.lay[l];
        cudaFree(ly.T_hi); cudaFree(ly.T_lo); cudaFree(ly.Zb); cudaFree(ly.Gr);
        cudaFree(ly.Zb_lo); cudaFree(ly.Gr_lo);
        cudaFree(ly.A0); cudaFree(ly.AD); cudaFree(ly.SSQ); cudaFree(ly.YD);
    }
    cudaFree(P.zl);
    cudaFree(P.Xf);
    cudaFree(P.red_a);
    cudaFree(P.red_g);
    cudaFree(P.red_a_lo);
    cudaFree(P.red_g_lo);
}

// Gram over rows: part[z][p][q] = sum_{rows in chunk z} X[row][p] Y[row][q].
// With X_lo and Y_lo (split-BF16 everywhere) the three products
// X_hi^T Y_hi + X_hi^T Y_lo + X_lo^T Y_hi are accumulated.  The row-chunk
// length comes from the tuning table, else from the wave model (measured
// first when the tuner may).
kfac_status_t gram(kfac_pinn_handle* h, cudaStream_t s, const CUtensorMap& X, const CUtensorMap& Y, int P, int Q,
                   int rows, int alg_rows, int sym, float* part, int& nz, const CUtensorMap* X_lo = nullptr,
                   const CUtensorMap* Y_lo = nullptr) {
    using C = tck::Cfg<tck::GRAM>;
    int p_tiles = (P + 127) / 128, q_tiles = (Q + C::BN - 1) / C::BN;
    int tiles = 0;
    for (int pb = 0; pb < p_tiles; pb++) tiles += q_tiles - (sym ? (pb * 128) / C::BN : 0);
    int max_chunks = (int)(MX(h)->gpart_region / ((size_t)P * Q));
    if (max_chunks > MAX_GRAM_CHUNKS) max_chunks = MAX_GRAM_CHUNKS;
    if (max_chunks < 1) return KFAC_BAD_ARG;
    const int split = (X_lo && Y_lo) ? 1 : 0;
    // every candidate needs at most max_chunks chunks of at most
    // GRAM_MAX_CHUNK_ROWS rows (the fewest chunks that fit when the workspace
    // cannot hold that many)
    Cands c;
    int want0 = (rows + GRAM_MAX_CHUNK_ROWS - 1) / GRAM_MAX_CHUNK_ROWS;
    if (want0 > max_chunks) want0 = max_chunks;
    if (want0 < 1) want0 = 1;
    for (int want = want0; want <= max_chunks; want++) {
        const int cl = round_up((rows + want - 1) / want, 64);
        const int cnt = (rows + cl - 1) / cl;
        if (cnt > max_chunks) continue;
        c.add(cl, wave_efficiency((long long)tiles * cnt, h->sm_count) * (double)rows / ((double)cnt * cl));
    }
    if (c.n == 0) return KFAC_BAD_ARG;

    Args a;
    memset(&a, 0, sizeof(a));
    a.a0 = X;
    a.b0 = Y;
    a.P = P;
    a.Q = Q;
    a.rows = rows;
    a.sym = sym;
    a.q_tiles = q_tiles;
    a.part = part;
    a.status = h->status;
    if (split) {
        a.a1 = *X_lo;
        a.b1 = *Y_lo;
        a.split_all = 1;
    }
    // the method's work: the n (n + 1) / 2 entries of a symmetric Gram (P x Q
    // otherwise) over the real rows, one product each; executed: whole tiles
    // over the padded rows, three products when split
    const double work = sym ? (double)P * (P + 1) * alg_rows : 2.0 * (double)P * Q * alg_rows;
    const double exec = 2.0 * (double)tiles * 128 * C::BN * rows * (split ? 3 : 1);
    auto launch = [&](int cl) {
        a.row_chunk = cl;
        return launch_engine<tck::GRAM>(h, s, a, dim3(tiles, (rows + cl - 1) / cl, 1), KFAC_KC_GRAM, work, exec);
    };

    int chunk = c.len[c.model];
    kfac_tune_entry_t key;
    memset(&key, 0, sizeof(key));
    key.kind = KFAC_TUNE_GRAM;
    key.P = P;
    key.Q = Q;
    key.K = rows;
    key.sym = sym;
    key.split = split;
    const int ti = tune_find(h, key);
    if (ti >= 0) {
        const int t = h->tune[ti].chunk;
        if (t >= 64 && t % 64 == 0 && t <= round_up(rows, 64) && (rows + t - 1) / t <= max_chunks) chunk = t;
    } else if (tune_may_measure(h, s)) {
        kfac_status_t st = tune_measure(h, s, key, c, launch, chunk);
        if (st) return st;
    }
    nz = (rows + chunk - 1) / chunk;
    return launch(chunk);
}

// ============================================================================
// Forward / backward of one pass
// ============================================================================
kfac_status_t convert_weights_into(kfac_pinn_handle* h, cudaStream_t s, const double* theta, MxWeights& w) {
    const int L = h->cfg.L;
    for (int l = 2; l <= L - 1; l++) {
        int hout = h->dims[l], hin = h->dims[l - 1];
        int hout_p = round_up(hout, 64), hin_p = round_up(hin, 64);
        KFAC_TRY(KL<k_convert_weights>(h, s, dim3(ceil_div_u(hin_p, 32), ceil_div_u(hout_p, 32)), 0,
                                       theta + h->woff[l - 1],
                                       hout, hin, hout_p, hin_p, w.W_hi[l - 1], w.W_lo[l - 1], w.Wt[l - 1],
                                       w.Wt_lo[l - 1], w.bias[l - 1]));
    }
    {
        const int h1 = h->dims[1], hp1 = round_up(h1, 64), d = h->dims[0];
        KFAC_TRY(KL<k_convert_first>(h, s, ceil_div_u((long long)(d + 1) * hp1, EW), 0, theta + h->woff[0], h1, hp1,
                                     d, w.W1f));
        if (w.W1Qf) {
            KFAC_TRY(KL<k_rotate_first>(h, s, ceil_div_u((long long)d * hp1, EW), 0, w.W1f, MX(h)->Qf, d, hp1,
                                        w.W1Qf));
        }
    }
    int hin = h->dims[L - 1], hin_p = round_up(hin, 64);
    KFAC_TRY(KL<k_convert_last>(h, s, ceil_div_u(hin_p + 1, EW), 0, theta + h->woff[L - 1], hin, hin_p, w.wL));
    return KFAC_OK;
}

kfac_status_t convert_weights(kfac_pinn_handle* h, cudaStream_t s, const double* theta) {
    return convert_weights_into(h, s, theta, MX(h)->w);
}

kfac_status_t forward_pass(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X, int N,
                           MxPass& P, BlockSel sel) {
    MxState* m = MX(h);
    const int L = h->cfg.L, d = h->dims[0], S = P.S;
    const int split = sel.split_all;     // split-BF16 on every row (else value / Laplacian / time rows only)
    {
        MxLayer& l1 = P.lay[0];
        long long cnt = (long long)P.N_pad * l1.hp;
        timer_begin(h, KFAC_KC_ELEMENTWISE, s);
        KFAC_TRY(KL<k_points_f32>(h, s, ceil_div_u((long long)P.N_pad * d, EW), 0, X, N, P.N_pad, d, P.Xf));
        KFAC_TRY(KL<k_layer1>(h, s, ceil_div_u(cnt / 4, EW), 0, m->w.W1f, m->w.W1Qf ? m->w.W1Qf : m->w.W1f, P.Xf, N,
                              P.N_pad, d, l1.h, l1.hp, S, h->chw32, (h->cfg.op == KFAC_OP_HEAT && S > 2) ? 1 : 0,
                              split, l1.T_hi, l1.T_lo, l1.A0, l1.AD, l1.SSQ));
        timer_end(h, KFAC_KC_ELEMENTWISE, s, 2.0 * (double)S * cnt + 16.0 * cnt);
    }
    for (int l = 2; l <= L - 1; l++) {
        MxLayer& in = P.lay[l - 2];
        MxLayer& out = P.lay[l - 1];
        Args a = base_args(h, P, N);
        a.split_all = split;
        a.a0 = in.kT_hi;
        a.a1 = in.kT_lo;
        const int jb = (out.hp + 127) / 128, pb = P.N_pad / 128;
        // CTA pairs over consecutive point blocks (grid: 2 x feature tiles,
        // point-block pairs; an odd count of point blocks leaves one CTA idle)
        const bool pair = h->cta_pairs != 0;
        const int pbx = pair ? pb + (pb & 1) : pb;
        a.b0 = pair ? m->w.kWp_hi[l - 1] : m->w.kW_hi[l - 1];
        a.b1 = pair ? m->w.kWp_lo[l - 1] : m->w.kW_lo[l - 1];
        a.k_steps = in.hp / 64;
        a.n_out = out.h;
        a.hp_out = out.hp;
        a.out_hi = out.T_hi;
        a.out_lo = out.T_lo;
        a.bias = m->w.bias[l - 1];
        a.A0 = out.A0;
        a.AD = out.AD;
        a.part = m->part;
        auto grid = [&](int z) { return pair ? dim3(2 * jb, pbx / 2, z) : dim3(jb, pb, z); };
        // per Taylor row block: the method's FLOPs (real sizes) and the executed
        // tensor FLOPs of one product over the padded tile
        const double alg = 2.0 * N * (double)out.h * in.h;
        const double fl = 2.0 * P.N_pad * (double)out.hp * in.hp;
        kfac_status_t st = launch_engine<tck::FWD_VALUE>(h, s, a, grid(1), KFAC_KC_LAYER_GEMM, alg, 3 * fl, pair);
        if (st) return st;
        if (S > 1) {
            const int tiles = S - 1;
            auto launch = [&](int len) {
                a.chunk_len = len;
                a.n_chunks = (tiles + len - 1) / len;
                return launch_engine<tck::FWD_TANLAP>(h, s, a, grid(a.n_chunks), KFAC_KC_LAYER_GEMM,
                                                      alg * (S - 1), fl * (a.split_all ? 3 * (S - 1) : S + 1), pair);
            };
            int len = 0;
            if ((st = tangent_chunk(h, s, KFAC_TUNE_FWD_TAN, split, P.N_pad, out.hp, in.hp, tiles, jb * pbx, launch,
                                    len)))
                return st;
            if ((st = launch(len))) return st;
            long long cnt = (long long)P.N_pad * out.hp;
            timer_begin(h, KFAC_KC_ELEMENTWISE, s);
            KFAC_TRY(KL<k_lap_finish>(h, s, ceil_div_u(cnt, EW), 0, m->part, a.n_chunks, N, P.N_pad, out.h, out.hp, S,
                                      out.A0, out.AD, out.SSQ, out.T_hi, out.T_lo, split));
            timer_end(h, KFAC_KC_ELEMENTWISE, s, (4.0 * a.n_chunks + 16.0) * cnt);
        }
    }
    MxLayer& last = P.lay[L - 2];
    long long threads = (long long)(sel.nsel ? sel.nsel : S) * P.N_pad * 32;
    timer_begin(h, KFAC_KC_ELEMENTWISE, s);
    KFAC_TRY(KL<k_last_fwd>(h, s, ceil_div_u(threads, EW), 0, last.T_hi, last.T_lo, m->w.wL, P.N_pad, S, last.hp, sel,
                            P.zl));
    timer_end(h, KFAC_KC_ELEMENTWISE, s, 0.0);
    return KFAC_OK;
}

kfac_status_t backward_pass(kfac_pinn_handle* h, cudaStream_t s, const double* r, int N, MxPass& P,
                            const float* seed = nullptr) {
    MxState* m = MX(h);
    const int L = h->cfg.L, S = P.S;
    {
        MxLayer& ly = P.lay[L - 2];
        long long cnt = (long long)P.N_pad * ly.hp;
        timer_begin(h, KFAC_KC_ELEMENTWISE, s);
        KFAC_TRY(KL<k_last_bwd>(h, s, ceil_div_u(cnt, EW), 0, m->w.wL, ly.T_hi, ly.A0, ly.AD, ly.SSQ, r, N, P.N_pad,
                                ly.h, ly.hp, S, h->chw32, (float)h->cT, (float)h->cD, seed, ly.Zb, ly.Gr,
                                ly.Zb_lo ? ly.T_lo : nullptr, ly.Zb_lo, ly.Gr_lo));
        timer_end(h, KFAC_KC_ELEMENTWISE, s, 6.0 * S * (double)cnt);
    }
    for (int l = L - 1; l >= 2; l--) {
        MxLayer& up = P.lay[l - 1];    // g^{(l)}
        MxLayer& dn = P.lay[l - 2];    // layer l-1 (output of the backward step)
        Args a = base_args(h, P, N);
        a.a0 = up.kZb;
        a.b0 = m->w.kWt[l - 1];
        if (a.split_all) {       // three products: G_hi W_hi + G_hi W_lo + G_lo W_hi
            a.a1 = up.kZb_lo;
            a.b1 = m->w.kWt_lo[l - 1];
            a.out_lo = dn.Zb_lo;
            a.out_gr_lo = dn.Gr_lo;
            a.ytan_lo = dn.T_lo;
        }
        a.k_steps = up.hp / 64;
        a.n_out = dn.h;
        a.hp_out = dn.hp;
        a.out_hi = dn.Zb;
        a.out_gr = dn.Gr;
        a.A0 = dn.A0;
        a.AD = dn.AD;
        a.SSQ = dn.SSQ;
        a.YD = dn.YD;
        a.part = m->part;
        a.ytan = dn.T_hi;
        a.r = r;
        const int jb = (dn.hp + 127) / 128, pb = P.N_pad / 128;
        const double alg = 2.0 * N * (double)up.h * dn.h;
        const double fl = 2.0 * P.N_pad * (double)up.hp * dn.hp * (a.split_all ? 3 : 1);
        kfac_status_t st;
        if (S > 1) {
            st = launch_engine<tck::BWD_LAP>(h, s, a, dim3(jb, pb, 1), KFAC_KC_ADJOINT_GEMM, alg, fl);
            if (st) return st;
            const int tiles = S - 2;
            auto launch = [&](int len) {
                a.chunk_len = len;
                a.n_chunks = (tiles + len - 1) / len;
                return launch_engine<tck::BWD_TAN>(h, s, a, dim3(jb, pb, a.n_chunks), KFAC_KC_ADJOINT_GEMM,
                                                   alg * (S - 2), fl * (S - 2));
            };
            int len = 0;
            if ((st = tangent_chunk(h, s, KFAC_TUNE_BWD_TAN, a.split_all, P.N_pad, dn.hp, up.hp, tiles, jb * pb,
                                    launch, len)))
                return st;
            if ((st = launch(len))) return st;
        }
        st = launch_engine<tck::BWD_VALUE>(h, s, a, dim3(jb, pb, 1), KFAC_KC_ADJOINT_GEMM, alg, fl);
        if (st) return st;
    }
    return KFAC_OK;
}

kfac_status_t factors_and_grad(kfac_pinn_handle* h, cudaStream_t s, const double* X, int N, const double* Xb,
                               int Nb) {
    MxState* m = MX(h);
    MxPass& I = m->in;
    MxPass& B = m->bd;
    const int L = h->cfg.L, d = h->dims[0], S = I.S;
    const double beta = h->cfg.beta;
    const bool reduce = (h->cfg.variant == KFAC_REDUCE);
    float* part_i = m->gpart;
    float* part_b = m->gpart + m->gpart_region;
    double* cs_i = m->cs;
    double* cs_b = m->cs + (m->hp_max + 8);
    kfac_status_t st;
    int zi = 0, zb = 0;
    const bool sa = is_split_all(h);     // split-BF16 everywhere: three-product Grams

    // ---- layer 1: closed-form A, gradient from the adjoints ---------------
    {
        int n1 = d + 1;
        KFAC_TRY(KL<k_factor_A1>(h, s, dim3(ceil_div_u(n1, 32), n1), 0, I.Xf, N, d, S, reduce, 0,
                                 h->fac[KFAC_A_INT][0], beta, h->status));
        KFAC_TRY(KL<k_factor_A1>(h, s, dim3(ceil_div_u(n1, 32), n1), 0, B.Xf, Nb, d, 1, 0, 1, h->fac[KFAC_A_BDY][0],
                                 beta, h->status));
        MxLayer& l1 = I.lay[0];
        KFAC_TRY(KL<k_grad_layer1>(h, s, dim3(ceil_div_u(l1.h, 32), d + 1), 0, l1.Gr, B.lay[0].Gr, I.Xf, B.Xf, N,
                                   I.N_pad, Nb, d, l1.h, l1.hp, S, 1.0 / N, 1.0 / Nb, h->grad + h->woff[0], m->gtan,
                                   l1.Gr_lo, B.lay[0].Gr_lo));
        if (m->gtan) {
            KFAC_TRY(KL<k_rotate_grad1>(h, s, ceil_div_u((long long)l1.h * d, EW), 0, m->gtan, m->Qf, l1.h, d,
                                        h->grad + h->woff[0]));
        }
    }
    // ---- hidden-layer output factors B_l, l = 1..L-1 -----------------------
    for (int l = 1; l <= L - 1; l++) {
        MxLayer& li = I.lay[l - 1];
        MxLayer& lb = B.lay[l - 1];
        if (reduce) {
            long long cnt = (long long)I.N_pad * li.hp;
            KFAC_TRY(KL<k_sum_over_s>(h, s, ceil_div_u(cnt, EW), 0, li.Zb, sa ? li.Zb_lo : nullptr, I.N_pad, S, li.hp,
                                      1.f, I.red_g, sa ? I.red_g_lo : nullptr));
            if ((st = gram(h, s, I.gRg[l - 1], I.gRg[l - 1], li.h, li.h, I.N_pad, N, 1, part_i, zi,
                           sa ? &I.gRg_lo[l - 1] : nullptr, sa ? &I.gRg_lo[l - 1] : nullptr)))
                return st;
        } else {
            if ((st = gram(h, s, li.gZb, li.gZb, li.h, li.h, I.rows, S * N, 1, part_i, zi, sa ? &li.gZb_lo : nullptr,
                           sa ? &li.gZb_lo : nullptr)))
                return st;
        }
        long long nn = (long long)li.h * li.h;
        KFAC_TRY(KL<k_factor_reduce>(h, s, ceil_div_u(nn, EW), 0, part_i, zi, li.h, 1, nullptr, 1.0 / N, 0.0, 0.0, 0,
                                     h->fac[KFAC_B_INT][l - 1], beta, h->status));
        if ((st = gram(h, s, lb.gZb, lb.gZb, lb.h, lb.h, B.rows, Nb, 1, part_b, zb, sa ? &lb.gZb_lo : nullptr,
                       sa ? &lb.gZb_lo : nullptr)))
            return st;
        KFAC_TRY(KL<k_factor_reduce>(h, s, ceil_div_u(nn, EW), 0, part_b, zb, lb.h, 1, nullptr, 1.0 / Nb, 0.0, 0.0, 0,
                                     h->fac[KFAC_B_BDY][l - 1], beta, h->status));
    }
    // ---- input factors A_l and gradients of layers 2..L ---------------------
    for (int l = 2; l <= L; l++) {
        MxLayer& ti = I.lay[l - 2];   // T^{(l-1)}
        MxLayer& tb = B.lay[l - 2];
        const int hin = ti.h;
        const long long nn = (long long)(hin + 1) * (hin + 1);
        // interior A_l
        if (reduce) {
            long long cnt = (long long)I.N_pad * ti.hp;
            KFAC_TRY(KL<k_sum_over_s>(h, s, ceil_div_u(cnt, EW), 0, ti.T_hi, sa ? ti.T_lo : nullptr, I.N_pad, S,
                                      ti.hp, 1.f / S, I.red_a, sa ? I.red_a_lo : nullptr));
            if ((st = gram(h, s, I.gRa[l - 2], I.gRa[l - 2], hin, hin, I.N_pad, N, 1, part_i, zi,
                           sa ? &I.gRa_lo[l - 2] : nullptr, sa ? &I.gRa_lo[l - 2] : nullptr)))
                return st;
            KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(hin, 32), 0, I.red_a, sa ? I.red_a_lo : nullptr, ti.hp, 0, N, hin,
                                  cs_i));
            KFAC_TRY(KL<k_factor_reduce>(h, s, ceil_div_u(nn, EW), 0, part_i, zi, hin, 1, cs_i, 1.0 / N,
                                         1.0 / ((double)N * S), 1.0 / ((double)S * S), 1, h->fac[KFAC_A_INT][l - 1],
                                         beta, h->status));
        } else {
            if ((st = gram(h, s, ti.gT, ti.gT, hin, hin, I.rows, S * N, 1, part_i, zi, sa ? &ti.gT_lo : nullptr,
                           sa ? &ti.gT_lo : nullptr)))
                return st;
            KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(hin, 32), 0, ti.T_hi, ti.T_lo, ti.hp, 0, N, hin, cs_i));
            double sc = 1.0 / ((double)N * S);
            KFAC_TRY(KL<k_factor_reduce>(h, s, ceil_div_u(nn, EW), 0, part_i, zi, hin, 1, cs_i, sc, sc, 1.0 / S, 1,
                                         h->fac[KFAC_A_INT][l - 1], beta, h->status));
        }
        // boundary A_l
        if ((st = gram(h, s, tb.gT, tb.gT, hin, hin, B.rows, Nb, 1, part_b, zb, sa ? &tb.gT_lo : nullptr,
                       sa ? &tb.gT_lo : nullptr)))
            return st;
        KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(hin, 32), 0, tb.T_hi, tb.T_lo, tb.hp, 0, Nb, hin, cs_b));
        KFAC_TRY(KL<k_factor_reduce>(h, s, ceil_div_u(nn, EW), 0, part_b, zb, hin, 1, cs_b, 1.0 / Nb, 1.0 / Nb, 1.0,
                                     1, h->fac[KFAC_A_BDY][l - 1], beta, h->status));
        // gradient of layer l
        if (l < L) {
            MxLayer& gi = I.lay[l - 1];
            MxLayer& gb = B.lay[l - 1];
            const int hout = gi.h;
            if ((st = gram(h, s, gi.gGr, ti.gT, hout, hin, I.rows, S * N, 0, part_i, zi, sa ? &gi.gGr_lo : nullptr,
                           sa ? &ti.gT_lo : nullptr)))
                return st;
            if ((st = gram(h, s, gb.gGr, tb.gT, hout, hin, B.rows, Nb, 0, part_b, zb, sa ? &gb.gGr_lo : nullptr,
                           sa ? &tb.gT_lo : nullptr)))
                return st;
            KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(hout, 32), 0, gi.Gr, gi.Gr_lo, gi.hp, 0, N, hout, cs_i));
            KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(hout, 32), 0, gb.Gr, gb.Gr_lo, gb.hp, 0, Nb, hout, cs_b));
            KFAC_TRY(KL<k_grad_reduce>(h, s, ceil_div_u((long long)hout * (hin + 1), EW), 0, part_i, zi, part_b, zb,
                                       hout, hin, cs_i, cs_b, 1.0 / N, 1.0 / Nb, h->grad + h->woff[l - 1]));
        } else {
            KFAC_TRY(KL<k_last_layer_terms>(h, s, ceil_div_u(hin + 1, 32), 0, ti.T_hi, ti.T_lo, tb.T_hi, tb.T_lo,
                                            h->in.r, h->bd.r, N, I.N_pad, Nb, B.N_pad, hin, ti.hp, S, h->cT, h->cD,
                                            reduce, h->grad + h->woff[L - 1], h->fac[KFAC_B_INT][L - 1],
                                            h->fac[KFAC_B_BDY][L - 1], beta, h->status, sa ? 1 : 0));
        }
    }
    return KFAC_OK;
}

}  // namespace

// ============================================================================
// Library-internal entry points
// ============================================================================
namespace {

// Device copies of one parameter vector in the layouts the kernels read.
kfac_status_t alloc_weights(kfac_pinn_handle* h, MxWeights& w) {
    const int L = h->cfg.L;
    kfac_status_t st;
    for (int l = 2; l <= L - 1; l++) {
        int hout_p = round_up(h->dims[l], 64), hin_p = round_up(h->dims[l - 1], 64);
        size_t e = (size_t)hout_p * hin_p;
        if ((st = dal(&w.W_hi[l - 1], e))) return st;
        if ((st = dal(&w.W_lo[l - 1], e))) return st;
        if ((st = dal(&w.Wt[l - 1], e))) return st;
        if ((st = dal(&w.bias[l - 1], (size_t)hout_p))) return st;
        bool ok = tc_make_tmap_2d(&w.kW_hi[l - 1], w.W_hi[l - 1], hin_p, hout_p, hin_p * 2, 64, 128) &&
                  tc_make_tmap_2d(&w.kW_lo[l - 1], w.W_lo[l - 1], hin_p, hout_p, hin_p * 2, 64, 128) &&
                  tc_make_tmap_2d(&w.kWp_hi[l - 1], w.W_hi[l - 1], hin_p, hout_p, hin_p * 2, 64, 64) &&
                  tc_make_tmap_2d(&w.kWp_lo[l - 1], w.W_lo[l - 1], hin_p, hout_p, hin_p * 2, 64, 64) &&
                  tc_make_tmap_2d(&w.kWt[l - 1], w.Wt[l - 1], hout_p, hin_p, hout_p * 2, 64, 128);
        if (!ok) return KFAC_CUDA_ERROR;
        if (is_split_all(h)) {
            if ((st = dal(&w.Wt_lo[l - 1], e))) return st;
            if (!tc_make_tmap_2d(&w.kWt_lo[l - 1], w.Wt_lo[l - 1], hout_p, hin_p, hout_p * 2, 64, 128))
                return KFAC_CUDA_ERROR;
        }
    }
    if ((st = dal(&w.wL, (size_t)round_up(h->dims[L - 1], 64) + 1))) return st;
    if ((st = dal(&w.W1f, (size_t)(h->dims[0] + 1) * round_up(h->dims[1], 64)))) return st;
    if (h->opQ && (st = dal(&w.W1Qf, (size_t)h->dims[0] * round_up(h->dims[1], 64)))) return st;
    return KFAC_OK;
}

void free_weights(MxWeights& w) {
    for (int l = 0; l < KFAC_MAX_LAYERS; l++) {
        cudaFree(w.W_hi[l]); cudaFree(w.W_lo[l]); cudaFree(w.Wt[l]); cudaFree(w.bias[l]);
        cudaFree(w.Wt_lo[l]);
    }
    cudaFree(w.wL);
    cudaFree(w.W1f);
    cudaFree(w.W1Qf);
}

}  // namespace

kfac_status_t tc_alloc(kfac_pinn_handle* h) {
    if (h->cfg.L < 2) return KFAC_BAD_ARG;   // the mixed path needs a hidden layer
    MxState* m = (MxState*)calloc(1, sizeof(MxState));
    if (!m) return KFAC_OOM;
    h->mx = m;
    kfac_status_t st;
    if ((st = alloc_pass(h, m->in, h->cfg.max_n_int, h->S))) return st;
    if ((st = alloc_pass(h, m->bd, h->cfg.max_n_bdy, 1))) return st;
    const int L = h->cfg.L;
    int hp_max = 64;
    for (int l = 0; l <= L; l++) hp_max = hp_max > round_up(h->dims[l], 64) ? hp_max : round_up(h->dims[l], 64);
    m->hp_max = hp_max;
    if ((st = alloc_weights(h, m->w))) return st;
    if (h->cfg.update == KFAC_UPDATE_AUTO) {
        if ((st = alloc_weights(h, m->dw))) return st;
        m->have_dw = true;
    }
    if (h->opQ) {
        const int d = h->dims[0];
        if ((st = dal(&m->Qf, (size_t)d * d))) return st;
        if ((st = dal(&m->gtan, (size_t)h->dims[1] * d))) return st;
        std::vector<double> q((size_t)d * d);
        std::vector<float> qf((size_t)d * d);
        if (cudaMemcpy(q.data(), h->opQ, sizeof(double) * d * d, cudaMemcpyDeviceToHost) != cudaSuccess)
            return KFAC_CUDA_ERROR;
        for (size_t i = 0; i < q.size(); i++) qf[i] = (float)q[i];
        if (cudaMemcpy(m->Qf, qf.data(), sizeof(float) * d * d, cudaMemcpyHostToDevice) != cudaSuccess)
            return KFAC_CUDA_ERROR;
    }
    if ((st = dal(&m->part, (size_t)MAX_CHUNKS * m->in.N_pad * hp_max))) return st;
    size_t maxPQ = (size_t)hp_max * hp_max;
    m->gpart_region = (size_t)MAX_GRAM_CHUNKS * maxPQ;
    if ((st = dal(&m->gpart, 2 * m->gpart_region))) return st;
    if ((st = dal(&m->cs, 2 * ((size_t)hp_max + 8)))) return st;
    if ((st = dal(&m->seed, (size_t)h->S * m->in.N_pad))) return st;
    if (cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->join, cudaEventDisableTiming) != cudaSuccess)
        return KFAC_CUDA_ERROR;
    return KFAC_OK;
}

void tc_free(kfac_pinn_handle* h) {
    MxState* m = MX(h);
    if (!m) return;
    free_pass(m->in);
    free_pass(m->bd);
    free_weights(m->w);
    if (m->have_dw) free_weights(m->dw);
    cudaFree(m->Qf);
    cudaFree(m->gtan);
    cudaFree(m->seed);
    cudaFree(m->part);
    cudaFree(m->gpart);
    cudaFree(m->cs);
    if (m->side) {
        cudaStreamSynchronize(m->side);
        cudaStreamDestroy(m->side);
    }
    if (m->fork) cudaEventDestroy(m->fork);
    if (m->join) cudaEventDestroy(m->join);
    free(m);
    h->mx = nullptr;
}

namespace {

// Input dimension from which a split-everywhere handle runs its line-search
// trial passes with plain BF16 tangent rows (see forward_and_residuals).
constexpr int TRIAL_BF16_TANGENTS_MIN_D = 32;

// Forward passes of both terms and their residuals into h->in.r / h->bd.r.
// trial: a line-search trial loss.  For d >= TRIAL_BF16_TANGENTS_MIN_D its
// forward pass keeps split-BF16 on the rows the residuals read through
// (value, second-order and heat time rows) and runs the tangent rows in plain
// BF16 also for a split-everywhere handle: the second-order row sums
// sigma'' a_i^2 over the d tangents, whose independent BF16 roundings average
// out like 1/sqrt(d) (trial losses within 1e-4 of FP64 at d = 100, 2e-4 at
// d = 5), and the tangent GEMMs are where that pass spends its time.  The
// curvature pass of the step (factors, gradient, direction) stays split on
// every row.
kfac_status_t forward_and_residuals(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X_int,
                                    int N_int, const double* f, const double* X_bdy, int N_bdy, const double* g,
                                    bool trial = false) {
    MxState* m = MX(h);
    kfac_status_t st;
    const int S = m->in.S;
    const int heat = h->cfg.op == KFAC_OP_HEAT;
    if ((st = convert_weights(h, s, theta))) return st;
    // boundary pass on the side stream: it fills the SMs the interior pass's
    // value GEMMs leave idle (its grids are N_bdy / 128 point blocks wide)
    BlockSel sb;
    sb.nsel = 1;
    sb.b[0] = 0;
    sb.b[1] = sb.b[2] = 0;
    sb.split_time = 0;
    const int split = (is_split_all(h) && !(trial && h->dims[0] >= TRIAL_BF16_TANGENTS_MIN_D)) ? 1 : 0;
    sb.split_all = split;
    KFAC_CUDA_TRY(cudaEventRecord(m->fork, s));
    KFAC_CUDA_TRY(cudaStreamWaitEvent(m->side, m->fork, 0));
    st = forward_pass(h, m->side, theta, X_bdy, N_bdy, m->bd, sb);
    if (st == KFAC_OK) {
        KFAC_TRY(KL<k_residual_mx>(h, m->side, ceil_div_u(N_bdy, EW), 0, m->bd.zl, g, h->bd.r, N_bdy, m->bd.N_pad, 1,
                                   0, h->cT, h->cD));
    }
    // the join is recorded even after an error, so that s never runs ahead of the side stream
    KFAC_CUDA_TRY(cudaEventRecord(m->join, m->side));
    if (st) {
        KFAC_CUDA_TRY(cudaStreamWaitEvent(s, m->join, 0));
        return st;
    }
    // interior: the residual needs the Laplacian row (and the time row for heat)
    BlockSel si;
    si.nsel = heat ? 2 : 1;
    si.b[0] = S - 1;
    si.b[1] = 1;
    si.b[2] = 0;
    si.split_time = heat;
    si.split_all = split;
    st = forward_pass(h, s, theta, X_int, N_int, m->in, si);
    if (st == KFAC_OK) {
        KFAC_TRY(KL<k_residual_mx>(h, s, ceil_div_u(N_int, EW), 0, m->in.zl, f, h->in.r, N_int, m->in.N_pad, S, 1,
                                   h->cT, h->cD));
    }
    KFAC_CUDA_TRY(cudaStreamWaitEvent(s, m->join, 0));
    return st;
}

}  // namespace

kfac_status_t tc_factors(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X_int, int N_int,
                         const double* f, const double* X_bdy, int N_bdy, const double* g, double* loss) {
    MxState* m = MX(h);
    kfac_status_t st;
    if ((st = forward_and_residuals(h, s, theta, X_int, N_int, f, X_bdy, N_bdy, g))) return st;
    if ((st = fp64_loss(h, s, N_int, N_bdy, loss))) return st;
    // the boundary adjoint beside the interior one (disjoint buffers)
    KFAC_CUDA_TRY(cudaEventRecord(m->fork, s));
    KFAC_CUDA_TRY(cudaStreamWaitEvent(m->side, m->fork, 0));
    const kfac_status_t sb = backward_pass(h, m->side, h->bd.r, N_bdy, m->bd);
    KFAC_CUDA_TRY(cudaEventRecord(m->join, m->side));
    st = backward_pass(h, s, h->in.r, N_int, m->in);
    KFAC_CUDA_TRY(cudaStreamWaitEvent(s, m->join, 0));
    if (sb) return sb;
    if (st) return st;
    return factors_and_grad(h, s, X_int, N_int, X_bdy, N_bdy);
}

kfac_status_t tc_eval_loss(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X_int, int N_int,
                           const double* f, const double* X_bdy, int N_bdy, const double* g, double* dst) {
    kfac_status_t st;
    if ((st = forward_and_residuals(h, s, theta, X_int, N_int, f, X_bdy, N_bdy, g, true))) return st;
    return fp64_loss_to(h, s, N_int, N_bdy, dst);
}

kfac_status_t tc_forward_laplacian(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X, int N,
                                   double* u, double* grad, double* lap) {
    MxState* m = MX(h);
    kfac_status_t st;
    if ((st = convert_weights(h, s, theta))) return st;
    BlockSel all;
    all.nsel = 0;
    all.b[0] = all.b[1] = all.b[2] = 0;
    all.split_time = (h->cfg.op == KFAC_OP_HEAT) ? 1 : 0;
    all.split_all = is_split_all(h) ? 1 : 0;
    if ((st = forward_pass(h, s, theta, X, N, m->in, all))) return st;
    KFAC_TRY(KL<k_extract_mx>(h, s, ceil_div_u(N, EW), 0, m->in.zl, N, m->in.N_pad, m->in.S, h->dims[0], m->Qf, u,
                              grad, lap));
    return KFAC_OK;
}

kfac_status_t tc_forward_laplacian_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X,
                                            int N, const double* du, const double* dgrad, const double* dlap,
                                            double* dtheta, double* dX, bool accumulate) {
    MxState* m = MX(h);
    MxPass& I = m->in;
    const int L = h->cfg.L, d = h->dims[0], S = I.S;
    const int heat = h->cfg.op == KFAC_OP_HEAT;
    kfac_status_t st;
    if ((st = convert_weights(h, s, theta))) return st;
    BlockSel all;
    all.nsel = 0;
    all.b[0] = all.b[1] = all.b[2] = 0;
    all.split_time = heat;
    all.split_all = is_split_all(h) ? 1 : 0;
    if ((st = forward_pass(h, s, theta, X, N, I, all))) return st;
    KFAC_TRY(KL<k_seed_mx>(h, s, ceil_div_u((long long)S * I.N_pad, EW), 0, m->seed, N, I.N_pad, S, m->Qf, du, dgrad,
                           dlap));
    if ((st = backward_pass(h, s, nullptr, N, I, m->seed))) return st;
    // gradient of every layer into the handle's gradient buffer, then into dtheta
    double* G = h->grad;
    float* part = m->gpart;
    double* cs = m->cs;
    int z = 0;
    {
        MxLayer& l1 = I.lay[0];
        KFAC_TRY(KL<k_grad_layer1>(h, s, dim3(ceil_div_u(l1.h, 32), d + 1), 0, l1.Gr, l1.Gr, I.Xf, I.Xf, N, I.N_pad,
                                   0, d, l1.h, l1.hp, S, 1.0, 0.0, G + h->woff[0], m->gtan, l1.Gr_lo, l1.Gr_lo));
        if (m->gtan) {
            KFAC_TRY(KL<k_rotate_grad1>(h, s, ceil_div_u((long long)l1.h * d, EW), 0, m->gtan, m->Qf, l1.h, d,
                                        G + h->woff[0]));
        }
    }
    for (int l = 2; l <= L - 1; l++) {
        MxLayer& ti = I.lay[l - 2];
        MxLayer& gi = I.lay[l - 1];
        const bool sa = is_split_all(h);
        if ((st = gram(h, s, gi.gGr, ti.gT, gi.h, ti.h, I.rows, S * N, 0, part, z, sa ? &gi.gGr_lo : nullptr,
                       sa ? &ti.gT_lo : nullptr)))
            return st;
        KFAC_TRY(KL<k_colsum>(h, s, ceil_div_u(gi.h, 32), 0, gi.Gr, sa ? gi.Gr_lo : nullptr, gi.hp, 0, N, gi.h, cs));
        KFAC_TRY(KL<k_grad_reduce>(h, s, ceil_div_u((long long)gi.h * (ti.h + 1), EW), 0, part, z, part, 0, gi.h,
                                   ti.h, cs, cs, 1.0, 0.0, G + h->woff[l - 1]));
    }
    {
        MxLayer& ti = I.lay[L - 2];
        KFAC_TRY(KL<k_last_grad_seeded>(h, s, ceil_div_u(ti.h + 1, 32), 0, ti.T_hi, ti.T_lo, m->seed, N, I.N_pad,
                                        ti.h, ti.hp, S, heat && S > 2, is_split_all(h) ? 1 : 0, G + h->woff[L - 1]));
    }
    KFAC_TRY(KL<k_copy_or_add>(h, s, ceil_div_u(h->D, EW), 0, dtheta, G, h->D, accumulate ? 1 : 0));
    if (dX) {
        const MxLayer& l1 = I.lay[0];
        KFAC_TRY(KL<k_dX_mx>(h, s, N, sizeof(float) * l1.hp, l1.Zb, is_split_all(h) ? l1.Zb_lo : nullptr, N, l1.hp,
                             l1.h, d, m->w.W1f, dX));
    }
    return KFAC_OK;
}

namespace {

// J_theta r . v for one pass whose forward activations at theta are held in P,
// with the direction v already converted into m->dw.
// J v of one pass (interior or boundary) for the direction converted into
// m->dw, from the pass's stored activations T^ and adjoints g (the step's
// curvature pass): jv[n] = sum_l sum_s g^{(l)}_{n,s}^T V~_l T^^{(l-1)}_{n,s}.
kfac_status_t jdot_pass(kfac_pinn_handle* h, cudaStream_t s, MxPass& P, int N, bool interior, double* jv) {
    MxState* m = MX(h);
    const int L = h->cfg.L, d = h->dims[0], S = P.S;
    const int heat = h->cfg.op == KFAC_OP_HEAT;
    const int split = is_split_all(h) ? 1 : 0;
    kfac_status_t st;
    // last layer (h_L = 1, g^{(L)}_{n,s} = c_s): jv = sum_s c_s (v_L . T^_{n,s} + [s = 0] b_v)
    {
        MxLayer& last = P.lay[L - 2];
        BlockSel sel;
        sel.b[0] = sel.b[1] = sel.b[2] = 0;
        sel.split_time = 0;
        sel.split_all = split;
        if (interior) {
            sel.nsel = heat ? 2 : 1;
            sel.b[0] = S - 1;
            sel.b[1] = 1;
            sel.split_time = heat;
        } else {
            sel.nsel = 1;
        }
        KFAC_TRY(KL<k_last_fwd>(h, s, ceil_div_u((long long)sel.nsel * P.N_pad * 32, EW), 0, last.T_hi, last.T_lo,
                                m->dw.wL, P.N_pad, S, last.hp, sel, P.zl));
        KFAC_TRY(KL<k_residual_jvp_mx>(h, s, ceil_div_u(N, EW), 0, P.zl, jv, N, P.N_pad, S, interior ? 1 : 0, h->cT,
                                       h->cD));
    }
    // hidden layers 2..L-1 on the tensor cores
    const long long part_cap = (long long)MAX_CHUNKS * m->in.N_pad * m->hp_max;
    for (int l = 2; l <= L - 1; l++) {
        MxLayer& in = P.lay[l - 2];    // T^{(l-1)}
        MxLayer& out = P.lay[l - 1];   // g^{(l)}
        Args a = base_args(h, P, N);
        a.a0 = in.kT_hi;
        a.a1 = in.kT_lo;
        a.b0 = m->dw.kW_hi[l - 1];
        a.b1 = m->dw.kW_lo[l - 1];
        a.k_steps = in.hp / 64;
        a.n_out = out.h;
        a.hp_out = out.hp;
        a.bias = m->dw.bias[l - 1];
        a.g_hi = out.Zb;
        a.g_lo = split ? out.Zb_lo : nullptr;
        a.part = m->part;
        const int jb = (out.hp + 127) / 128, pb = P.N_pad / 128;
        choose_chunks(S, jb * pb, h->sm_count, a.chunk_len, a.n_chunks);
        const int slots = a.n_chunks * jb * 2;
        if ((long long)slots * P.N_pad > part_cap) return KFAC_BAD_ARG;
        // three products on split rows (every row when split everywhere; the
        // value, second-order and time rows otherwise), one on plain BF16 rows
        const int split_rows = split ? S : (S == 1 ? 1 : (heat && S > 2 ? 3 : 2));
        const double alg = 2.0 * N * (double)S * out.h * in.h;
        const double fl = 2.0 * P.N_pad * (double)out.hp * in.hp;
        if ((st = launch_engine<tck::JDOT>(h, s, a, dim3(jb, pb, a.n_chunks), KFAC_KC_LAYER_GEMM, alg,
                                           fl * (S + 2 * split_rows))))
            return st;
        KFAC_TRY(KL<k_jdot_reduce>(h, s, ceil_div_u(N, EW), 0, m->part, slots, N, P.N_pad, jv));
    }
    // first layer
    {
        MxLayer& l1 = P.lay[0];
        const float* V1t = m->dw.W1Qf ? m->dw.W1Qf : m->dw.W1f;
        KFAC_TRY(KL<k_jdot_layer1>(h, s, N, 0, m->dw.W1f, V1t, P.Xf, l1.Zb, split ? l1.Zb_lo : nullptr, N, P.N_pad, d,
                                   l1.hp, S, jv));
    }
    return KFAC_OK;
}

}  // namespace

namespace {
// Self-check of the engine's mbarrier bound: a barrier expecting one arrival
// that never comes, waited on with limit_ns (kfac_pinn_check_wait_timeout).
__global__ void k_check_mbar_wait(int* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit_ns)) latch_status(status, KFAC_TIMEOUT);
}
}  // namespace

kfac_status_t tc_check_wait(kfac_pinn_handle* h, cudaStream_t s, uint64_t limit_ns) {
    k_check_mbar_wait<<<1, 32, 0, s>>>(h->status, limit_ns);
    KFAC_LAUNCH_CHECK(h);
    KFAC_CUDA_TRY(cudaStreamSynchronize(s));
    return KFAC_OK;
}

kfac_status_t tc_residual_jvp(kfac_pinn_handle* h, cudaStream_t s, const double* v, int N_int, int N_bdy,
                              double* jv_int, double* jv_bdy) {
    MxState* m = MX(h);
    if (!m->have_dw) return KFAC_BAD_ARG;
    kfac_status_t st;
    if ((st = convert_weights_into(h, s, v, m->dw))) return st;
    if ((st = jdot_pass(h, s, m->in, N_int, true, jv_int))) return st;
    return jdot_pass(h, s, m->bd, N_bdy, false, jv_bdy);
}
